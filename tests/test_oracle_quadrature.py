"""Pins for the oracle's contour quadrature and rational filter.

The guide does not print the quadrature formula; these tests pin the
oracle's reading (Gauss-Legendre in the angle of a circle through Emin and
Emax, weights from the residue theorem) against facts fixed by mathematics:
library Gauss-Legendre, exact polynomial integration, and the values of the
exact spectral projector's filter (1 inside, 1/2 on the circle, 0 outside)."""
import numpy as np
import pytest

import oracle

GL_ALLOWED = list(range(1, 21)) + [24, 32, 40, 48, 56]


@pytest.mark.parametrize("ne", GL_ALLOWED)
def test_gauss_legendre_matches_numpy(ne):
    x, w = oracle.gauss_legendre(ne)
    xr, wr = np.polynomial.legendre.leggauss(ne)
    assert np.allclose(x, xr, atol=1e-14, rtol=0)
    assert np.allclose(w, wr, atol=1e-14, rtol=0)


@pytest.mark.parametrize("ne", [1, 2, 5, 8, 16, 24])
def test_gauss_legendre_exact_on_polynomials(ne):
    x, w = oracle.gauss_legendre(ne)
    for k in range(2 * ne):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x**k) - exact) < 1e-13


@pytest.mark.parametrize("qtype", [0, 1])
@pytest.mark.parametrize("ne", [1, 3, 8, 16, 20, 56])
@pytest.mark.parametrize("emin,emax", [(-5.0, 5.0), (0.5, 1.0), (-2.3e-3, 2.3e-3), (0.0, 0.04)])
def test_filter_exact_values(ne, qtype, emin, emax):
    """For a circle the filter equals 1 at the centre and 1/2 at both ends,
    for any node count (Re[e^{it}/(e^{it}-1)] = 1/2)."""
    r0 = 0.5 * (emin + emax)
    f = oracle.rational(emin, emax, ne, np.array([r0, emin, emax]), qtype=qtype)
    assert abs(f[0] - 1.0) < 1e-13
    # at the ends, node real parts r0 + R cos(theta) cancel near cos = -1/+1,
    # so the rounding error grows with ne: tolerance 1e-15 * ne^2
    tol = max(1e-13, 1e-15 * ne * ne)
    assert abs(f[1] - 0.5) < tol
    assert abs(f[2] - 0.5) < tol


@pytest.mark.parametrize("ne", [8, 16])
def test_nodes_on_upper_half_circle(ne):
    emin, emax = -1.5, 4.0
    z, w = oracle.contour(emin, emax, ne)
    r0, R = 0.5 * (emin + emax), 0.5 * (emax - emin)
    assert np.allclose(np.abs(z - r0), R, rtol=0, atol=1e-14)
    assert np.all(z.imag > 0)
    # nodes run from the Emin side to the Emax side
    assert np.all(np.diff(z.real) > 0)
    # weights are (1/2) omega_e (z_e - r0): real parts sum to 0 by symmetry,
    # |w_e| / R sums to 1 (= sum omega / 2)
    assert abs(np.sum(np.abs(w)) / R - 1.0) < 1e-14


def test_filter_converges_to_projector():
    """With many nodes the filter tends to the exact indicator of the
    interval (residue theorem), away from the ends."""
    emin, emax = 1.0, 3.0
    inside = np.linspace(1.2, 2.8, 9)
    outside = np.concatenate([np.linspace(-10, 0.6, 7), np.linspace(3.4, 20, 7)])
    f_in = oracle.rational(emin, emax, 56, inside)
    f_out = oracle.rational(emin, emax, 56, outside)
    assert np.max(np.abs(f_in - 1.0)) < 1e-8
    assert np.max(np.abs(f_out)) < 1e-8


def test_filter_symmetry_and_decay():
    emin, emax = -1.0, 1.0
    t = np.linspace(0.0, 5.0, 41)
    f_plus = oracle.rational(emin, emax, 8, t)
    f_minus = oracle.rational(emin, emax, 8, -t)
    assert np.allclose(f_plus, f_minus, rtol=0, atol=1e-14)
    far = np.abs(oracle.rational(emin, emax, 8, np.array([3.0, 10.0, 100.0])))
    assert far[0] < 1e-5 and far[1] < 1e-8 and far[2] < 1e-12
    assert far[0] > far[1] > far[2]


def test_trapezoid_weights_equal():
    z, w = oracle.contour(0.0, 2.0, 6, qtype=1)
    assert np.allclose(np.abs(w), np.abs(w[0]), rtol=1e-15)


def test_ellipse_ratio_filter_at_centre():
    """For an ellipse (fpm(18) != 100) the centre value is 1 only up to the
    quadrature error, and converges to 1 as nodes are added."""
    f8 = oracle.rational(0.0, 2.0, 8, np.array([1.0]), ratio=50)[0]
    f56 = oracle.rational(0.0, 2.0, 56, np.array([1.0]), ratio=50)[0]
    assert abs(f56 - 1.0) < 1e-10
    assert abs(f56 - 1.0) < abs(f8 - 1.0) + 1e-15
