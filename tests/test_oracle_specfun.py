"""Pins of the oracle's special functions against independent libraries
(scipy.special, sympy exact 3j, mpmath) and identities."""
import math

import mpmath
import numpy as np
import pytest
import scipy.special as sp
from sympy.physics.wigner import wigner_3j

from oracle.specfun import legendre_norm, riccati_psi_all, sph_h1_all, sph_jn_all, sph_yn_all, wigner3j


@pytest.mark.parametrize("x", [1e-3, 0.3, 1.0, math.pi, 2 * math.pi, 4.493409457909064, 7.7, 25.0, 60.0])
def test_spherical_bessel_vs_scipy(x):
    lmax = 16
    j = sph_jn_all(lmax, x).real
    y = sph_yn_all(lmax, x).real
    jr = sp.spherical_jn(np.arange(lmax + 1), x)
    yr = sp.spherical_yn(np.arange(lmax + 1), x)
    scale = np.maximum(np.abs(jr), 1e-3 * np.max(np.abs(jr)))  # absolute near zeros
    assert np.all(np.abs(j - jr) <= 1e-12 * scale + 1e-300)
    assert np.all(np.abs(y - yr) <= 1e-12 * np.abs(yr))


def test_spherical_bessel_complex_vs_mpmath():
    z = 2.0 * 1.3 + 0.4j
    j = sph_jn_all(8, z)
    for l in range(9):
        ref = complex(mpmath.sqrt(mpmath.pi / (2 * z)) * mpmath.besselj(l + 0.5, z))
        assert abs(j[l] - ref) <= 1e-12 * abs(ref)


def test_hankel_wronskian():
    # j_l y_{l-1} - j_{l-1} y_l = 1/x^2  (A&S 10.1.6)
    for x in [0.7, 3.14159, 12.0]:
        h = sph_h1_all(12, x)
        j, y = h.real, h.imag
        for l in range(1, 13):
            assert abs(j[l] * y[l - 1] - j[l - 1] * y[l] - 1 / x ** 2) < 1e-12 / x ** 2


def test_riccati_derivative_fd():
    z = 1.7
    psi, dpsi = riccati_psi_all(6, z)
    h = 1e-6
    psip, _ = riccati_psi_all(6, z + h)
    psim, _ = riccati_psi_all(6, z - h)
    assert np.allclose(dpsi, (psip - psim) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("theta", [0.0, 0.3, math.pi / 2, 2.5, math.pi])
def test_legendre_normalised_vs_mpmath(theta):
    lmax = 10
    P, pi, tau = legendre_norm(lmax, theta)
    c = math.cos(theta)
    for l in range(lmax + 1):
        for m in range(l + 1):
            # mpmath.legenp includes the Condon-Shortley phase (-1)^m for |x| < 1
            ref = float(mpmath.legenp(l, m, c, type=2)) * (-1) ** m if abs(c) < 1 else (1.0 if m == 0 and c > 0 else (float((-1) ** l) if m == 0 else 0.0))
            ref *= math.sqrt((2 * l + 1) / 2 * math.factorial(l - m) / math.factorial(l + m))
            assert abs(P[l, m] - ref) < 1e-12


def test_legendre_orthonormal():
    # int_{-1}^{1} Pbar_l^m Pbar_l'^m dx = delta_ll'  (the normalisation of App. I-A)
    xg, wg = np.polynomial.legendre.leggauss(40)
    tabs = [legendre_norm(8, math.acos(x))[0] for x in xg]
    for m in range(0, 5):
        for l in range(m, 9):
            for lp in range(m, 9):
                v = sum(w * t[l, m] * t[lp, m] for w, t in zip(wg, tabs))
                assert abs(v - (1.0 if l == lp else 0.0)) < 1e-12


@pytest.mark.parametrize("theta", [0.2, 1.0, 2.9])
def test_pi_tau_fd(theta):
    P, pi, tau = legendre_norm(8, theta)
    h = 1e-6
    Pp = legendre_norm(8, theta + h)[0]
    Pm = legendre_norm(8, theta - h)[0]
    assert np.allclose(tau, (Pp - Pm) / (2 * h), atol=1e-7)
    for l in range(1, 9):
        for m in range(1, l + 1):
            assert abs(pi[l, m] - P[l, m] / math.sin(theta)) < 1e-12


def test_wigner3j_vs_sympy():
    rng = np.random.default_rng(5)
    for _ in range(300):
        j1, j2 = rng.integers(0, 9, size=2)
        j3 = rng.integers(abs(j1 - j2), j1 + j2 + 1)
        m1 = rng.integers(-j1, j1 + 1)
        m2 = rng.integers(-j2, j2 + 1)
        ref = float(wigner_3j(int(j1), int(j2), int(j3), int(m1), int(m2), int(-m1 - m2)))
        assert abs(wigner3j(int(j1), int(j2), int(j3), int(m1), int(m2), int(-m1 - m2)) - ref) < 1e-14


def test_wigner3j_orthogonality():
    # sum_{m1,m2} (j1 j2 j3; m1 m2 m3)(j1 j2 j3'; m1 m2 m3') = delta/(2j3+1)
    j1, j2 = 3, 4
    for j3 in range(1, 8):
        for j3p in range(1, 8):
            for m3 in range(-min(j3, j3p), min(j3, j3p) + 1):
                s = sum(wigner3j(j1, j2, j3, m1, -m1 - m3, m3) * wigner3j(j1, j2, j3p, m1, -m1 - m3, m3)
                        for m1 in range(-j1, j1 + 1))
                assert abs(s - (1 / (2 * j3 + 1) if j3 == j3p else 0)) < 1e-14
