"""Comparison helpers for the GPU parity tests (test code only).

Acceptance gates (the readings recorded in the design notes):
  * eigenvalues: |l_gpu - l_ref| <= TOL_E * max(|l_ref|, alpha),
    alpha = max(|Emin|, |Emax|) (the scale the guide's residual uses);
  * per-pair residual ||A x - l B x||_2 / (||A||_1 ||x||_2) <= TOL_R;
  * the eigenvectors of simple eigenvalues agree up to a unit phase, checked
    through |x_gpu^H B x_ref| ~= 1 (both B-normalised).
"""
import numpy as np

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
