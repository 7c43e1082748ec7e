"""Comparison helpers for the GPU parity tests (test code only).

Acceptance gates (the readings recorded in the design notes):
  * eigenvalues: |l_gpu - l_ref| <= TOL_E * max(|l_ref|, alpha),
    alpha = max(|Emin|, |Emax|) (the scale the guide's residual uses);
  * per-pair residual ||A x - l B x||_2 / (||A||_1 ||x||_2) <= TOL_R;
  * the eigenvectors of simple eigenvalues agree up to a unit phase, checked
    through |x_gpu^H B x_ref| ~= 1 (both B-normalised).
"""
import numpy as np

from paper_1203_4031_gb300 import workloads as W

TOL_E = 1e-10
TOL_R = 1e-10


def alpha(emin, emax):
    return max(abs(emin), abs(emax))


def residuals(A, B, X, E):
    """||A x - l B x||_2 / (||A||_1 ||x||_2) per column (FP64, numpy)."""
    AX = A @ X
    BX = X if B is None else B @ X
    R = AX - BX * E[None, :]
    nA = np.linalg.norm(A, 1)
    return np.linalg.norm(R, axis=0) / (nA * np.linalg.norm(X, axis=0))


def b_orth_error(B, X):
    BX = X if B is None else B @ X
    G = X.conj().T @ BX
    return np.max(np.abs(G - np.eye(X.shape[1])))


def compare_eigs(E_gpu, E_ref, emin, emax, tol=TOL_E):
    E_gpu = np.asarray(E_gpu)
    E_ref = np.asarray(E_ref)
    assert E_gpu.shape == E_ref.shape, (E_gpu.shape, E_ref.shape)
    scale = np.maximum(np.abs(E_ref), alpha(emin, emax))
    err = np.abs(E_gpu - E_ref) / scale
    return float(err.max()) if err.size else 0.0


def vector_alignment(B, Xg, Xr, E, gap_tol=1e-6):
    """min over simple eigenvalues of |x_gpu^H B x_ref| (1 = same vector)."""
    BX = Xr if B is None else B @ Xr
    ov = np.abs(np.sum(Xg.conj() * BX, axis=0))
    simple = np.ones(len(E), dtype=bool)
    d = np.diff(E)
    close = np.abs(d) < gap_tol * max(1.0, np.abs(E).max())
    simple[:-1] &= ~close
    simple[1:] &= ~close
    return float(ov[simple].min()) if simple.any() else 1.0


# ---- stochastic count (fpm(14)=2) inputs: probes and a gapped pencil ----
SEED = 0x3C6EF372FE94F82B   # the documented seed of generated subspaces / probes


def rademacher(n, m, seed=SEED):
    """+1 / -1 by the top bit of SplitMix64 at the column-major index."""
    bits = W.splitmix64(seed, np.arange(n * m, dtype=np.uint64)) >> np.uint64(63)
    return np.where(bits.reshape(m, n).T == 1, -1.0, 1.0)


def gapped_pencil(n, inside, herm, gen, seed):
    """A, B with a B-orthonormal eigenbasis V and eigenvalues: `inside` of
    them in [-0.5, 0.5], the rest with |lambda| in [2, 6]; interval [-1, 1]."""
    r = np.random.default_rng(seed)
    cplx = (lambda s: r.standard_normal(s) + 1j * r.standard_normal(s)) if herm else r.standard_normal
    U, _ = np.linalg.qr(cplx((n, n)))
    lam = np.concatenate([r.uniform(-0.5, 0.5, inside),
                          r.choice([-1.0, 1.0], n - inside) * r.uniform(2.0, 6.0, n - inside)])
    if gen:
        G = cplx((n, n))
        B = G @ G.conj().T / n + np.eye(n)
        L = np.linalg.cholesky(B)
        V = np.linalg.solve(L.conj().T, U)            # V^H B V = I
        A = B @ V @ np.diag(lam) @ V.conj().T @ B     # A V = B V diag(lam)
    else:
        B, V = None, U
        A = U @ np.diag(lam) @ U.conj().T
    A = np.asfortranarray(0.5 * (A + A.conj().T))
    if B is not None:
        B = np.asfortranarray(0.5 * (B + B.conj().T))
    return A, B, V, lam
