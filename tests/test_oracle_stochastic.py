"""Pins for the oracle's stochastic eigenvalue count (fpm(14)=2, the guide's
"Stochastic estimate" section; the estimator of Di Napoli, Polizzi & Saad).

One contour filters the probe block Y into Q = f(B^-1 A) Y; res(j) is the mean
of Re(y_i^H q_i) over the first j probes and M is res(M0) rounded.  The pins
use no quadrature: with a spectrum kept well away from the interval ends and
48 Gauss nodes, f is the indicator of the interval to rounding level, so
f(B^-1 A) is the spectral projector V_in V_in^H B built from a known
B-orthonormal eigenbasis, and every probe's quadratic form follows from it."""
import numpy as np
import pytest

import oracle

from feast_check import gapped_pencil, rademacher

def estimate(A, B, m0, herm, probes=None, ne=48, emin=-1.0, emax=1.0):
    fpm = oracle.feastinit()
    fpm[1] = ne
    fpm[13] = 2
    if probes is not None:
        fpm[4] = 1
    return oracle.feast(A, B, emin, emax, m0, fpm=fpm, X0=probes, hermitian=herm)


@pytest.mark.parametrize("herm,gen", [(False, False), (False, True), (True, False), (True, True)])
def test_running_mean_of_probe_quadratic_forms(herm, gen):
    n, inside, m0 = 72, 9, 11
    A, B, V, lam = gapped_pencil(n, inside, herm, gen, seed=5 + 2 * herm + gen)
    Y = rademacher(n, m0, seed=77)
    r = estimate(A, B, m0, herm, probes=Y)
    assert r["info"] == 5 and r["loop"] == 0
    sel = np.abs(lam) <= 0.5
    Vin = V[:, sel]
    Bm = np.eye(n) if B is None else B
    t = np.real(np.einsum("ij,ij->j", (Vin.conj().T @ Y).conj(), Vin.conj().T @ (Bm @ Y)))
    expect = np.cumsum(t) / np.arange(1, m0 + 1)
    assert np.allclose(r["res"], expect, rtol=0, atol=1e-10 * max(1.0, np.abs(t).max()))
    assert r["M"] == max(0, int(np.floor(expect[-1] + 0.5)))
    assert np.array_equal(r["X"], Y)                  # X returns the probes
    assert not np.any(r["E"])


def test_diagonal_matrix_gives_the_count_on_every_probe():
    """For diagonal A and B = I, y^T f(A) y = sum_i y_i^2 f(lambda_i) =
    sum_i f(lambda_i) for any +-1 probe: each running mean is the count."""
    r = np.random.default_rng(9)
    lam = np.concatenate([r.uniform(-0.5, 0.5, 13), r.uniform(2.0, 5.0, 40), -r.uniform(2.0, 5.0, 27)])
    A = np.diag(r.permutation(lam))
    res = estimate(A, None, 17, False)
    assert res["info"] == 5 and res["M"] == 13
    assert np.allclose(res["res"], 13.0, rtol=0, atol=1e-9)


@pytest.mark.parametrize("herm", [False, True])
def test_generated_probes_are_splitmix_rademacher(herm):
    n, m0 = 50, 6
    A, B, V, lam = gapped_pencil(n, 5, herm, True, seed=21 + herm)
    r = estimate(A, B, m0, herm)
    assert r["info"] == 5
    assert np.array_equal(r["X"], rademacher(n, m0))
    again = estimate(A, B, m0, herm, probes=rademacher(n, m0))
    assert np.array_equal(r["res"], again["res"])


def test_dense_estimate_lies_within_its_statistical_spread():
    """Dense real symmetric A, B = I: per probe Var(y^T P y) =
    2 (||P||_F^2 - sum_i P_ii^2) for a symmetric P and +-1 entries; with the
    default 8 nodes the mean over M0 probes lies within 5 standard errors of
    trace f(A), itself within 0.1 of the count for this gapped spectrum."""
    n, inside, m0 = 400, 25, 160
    A, B, V, lam = gapped_pencil(n, inside, False, False, seed=33)
    r = estimate(A, None, m0, False, ne=8)
    assert r["info"] == 5
    P = V[:, np.abs(lam) <= 0.5]
    P = P @ P.T
    sd = np.sqrt(2.0 * (np.sum(P * P) - np.sum(np.diag(P) ** 2)) / m0)
    assert abs(r["res"][-1] - inside) < 5 * sd + 0.1
    assert abs(r["M"] - inside) <= int(np.ceil(5 * sd + 0.1))


def test_empty_interval_estimates_zero():
    A = np.diag(np.r_[np.linspace(2.0, 5.0, 20), -np.linspace(2.0, 5.0, 20)])
    r = estimate(A, None, 8, False)
    assert r["info"] == 5 and r["M"] == 0
    assert np.all(np.abs(r["res"]) < 1e-9)


def test_complex_probes_use_the_conjugate_transpose():
    """Caller probes with unit-modulus complex entries (E[|y_i|^2] = 1, so the
    mean still estimates the trace): the form is y^H P y, not y^T P y."""
    n, inside, m0 = 64, 7, 9
    A, B, V, lam = gapped_pencil(n, inside, True, True, seed=41)
    r = np.random.default_rng(4)
    Y = np.exp(2j * np.pi * r.uniform(size=(n, m0)))
    out = estimate(A, B, m0, True, probes=Y)
    Vin = V[:, np.abs(lam) <= 0.5]
    t = np.real(np.einsum("ij,ij->j", (Vin.conj().T @ Y).conj(), Vin.conj().T @ (B @ Y)))
    assert np.allclose(out["res"], np.cumsum(t) / np.arange(1, m0 + 1), rtol=0, atol=1e-9)
