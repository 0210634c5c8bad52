"""Pins of the wave functions (App. I-A) and of the sphere T-matrix (Mie, the
sphere case of App. I-B)."""
import math

import mpmath
import numpy as np
import pytest
import scipy.special as sp

from oracle import mie, vswf
from oracle_pins import K0, mie_dipole_pattern_ratio, mie_extinction_error


def _curl(f, x, h=1e-5):
    J = np.zeros((3, 3) + f(x).shape[:-1], dtype=np.complex128)  # J[a, b] = d f_b / d x_a
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        J[a] = np.moveaxis((f(x + e) - f(x - e)) / (2 * h), -1, 0)
    return np.stack([J[1, 2] - J[2, 1], J[2, 0] - J[0, 2], J[0, 1] - J[1, 0]], axis=-1)


def _div(f, x, h=1e-5):
    s = 0
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        s = s + (f(x + e)[..., a] - f(x - e)[..., a]) / (2 * h)
    return s


def _scalar_wave(l, m, x, regular):
    """phi_lm / Rphi_lm written from the definition with scipy's functions."""
    r = np.linalg.norm(x)
    th = math.acos(x[2] / r)
    ph = math.atan2(x[1], x[0])
    z = sp.spherical_jn(l, K0 * r) + (0 if regular else 1j * sp.spherical_yn(l, K0 * r))
    am = abs(m)
    pbar = (-1) ** am * sp.lpmv(am, l, math.cos(th)) * math.sqrt((2 * l + 1) / 2 * math.factorial(l - am) / math.factorial(l + am))
    return z * pbar * np.exp(1j * m * ph)


@pytest.mark.parametrize("regular", [False, True])
def test_vswf_definition_by_finite_differences(regular):
    """Phi_{lm0} = grad(phi_lm) x r / sqrt(2l(l+1)); Phi_{lm1} = curl(Phi_{lm0})/k;
    curl Phi_{lm1} = k Phi_{lm0}; div Phi = 0."""
    nmax = 3
    L = nmax * (nmax + 2)
    rng = np.random.default_rng(3)
    f = lambda y: vswf.vswf(nmax, K0, y, regular=regular)
    for _ in range(3):
        x = rng.normal(size=3) * 0.4
        V = f(x)
        for (l, m) in vswf.lm_list(nmax):
            n = vswf.n_index(l, m)
            h = 1e-6
            grad = np.array([(_scalar_wave(l, m, x + h * e, regular) - _scalar_wave(l, m, x - h * e, regular)) / (2 * h)
                             for e in np.eye(3)])
            M = np.cross(grad, x) / math.sqrt(2 * l * (l + 1))
            assert np.allclose(V[n], M, atol=2e-6 * (1 + np.max(np.abs(M))))
        C = _curl(f, x)
        scale = np.max(np.abs(V))
        assert np.max(np.abs(C[:L] / K0 - V[L:])) < 1e-6 * scale
        assert np.max(np.abs(C[L:] / K0 - V[:L])) < 1e-6 * scale
        assert np.max(np.abs(_div(f, x))) < 1e-6 * K0 * scale


def test_mie_lossless_unitarity():
    """For a lossless sphere every mode satisfies |1 + 2t| = 1 (Re t = -|t|^2)."""
    for r in [0.05, 0.12, 0.2, 0.24]:
        t = mie.tmatrix_diag(6, K0, r, 2.0)
        assert np.max(np.abs(np.abs(1 + 2 * t) - 1)) < 1e-13


def test_mie_rayleigh_limit():
    """a_1 -> -(2i/3) x^3 (m^2-1)/(m^2+2) as x -> 0 (Bohren & Huffman 5.2)."""
    m = 2.0
    for x in [1e-3, 3e-3]:
        a, b = mie.mie_ab(3, K0, x / K0, m)
        ref = -2j / 3 * x ** 3 * (m * m - 1) / (m * m + 2)
        assert abs(a[1] - ref) < 1e-4 * abs(ref) + 1e-20
        assert abs(b[1]) < 1e-3 * abs(a[1])  # magnetic dipole is O(x^5)


def test_mie_vs_mpmath_high_precision():
    """Independent evaluation of the Bohren-Huffman coefficients with mpmath at
    40 digits (half-integer Bessel functions)."""
    mpmath.mp.dps = 40
    x = mpmath.mpf(2) * mpmath.pi * mpmath.mpf("0.23")
    m = mpmath.mpc(2.0, 0.05)
    psi = lambda l, z: z * mpmath.sqrt(mpmath.pi / (2 * z)) * mpmath.besselj(l + mpmath.mpf(1) / 2, z)
    xi = lambda l, z: z * mpmath.sqrt(mpmath.pi / (2 * z)) * (mpmath.besselj(l + mpmath.mpf(1) / 2, z) + 1j * mpmath.bessely(l + mpmath.mpf(1) / 2, z))
    dpsi = lambda l, z: mpmath.diff(lambda u: psi(l, u), z)
    dxi = lambda l, z: mpmath.diff(lambda u: xi(l, u), z)
    a, b = mie.mie_ab(5, K0, 0.23, complex(m))
    for l in range(1, 6):
        am = (m * psi(l, m * x) * dpsi(l, x) - psi(l, x) * dpsi(l, m * x)) / (m * psi(l, m * x) * dxi(l, x) - xi(l, x) * dpsi(l, m * x))
        bm = (psi(l, m * x) * dpsi(l, x) - m * psi(l, x) * dpsi(l, m * x)) / (psi(l, m * x) * dxi(l, x) - m * xi(l, x) * dpsi(l, m * x))
        assert abs(a[l] - complex(am)) < 1e-12 * abs(complex(am))
        assert abs(b[l] - complex(bm)) < 1e-12 * abs(complex(bm))
    mpmath.mp.dps = 15


def test_mie_extinction_and_far_field_power():
    """C_ext from the coefficients equals B-H's C_ext; the far-field quadrature of
    the oracle's field equals C_sca; for real m, C_ext = C_sca."""
    assert mie_extinction_error(1.3, 2.0) < 1e-12
    assert mie_extinction_error(0.6, 1.5) < 1e-12


def test_mie_electric_dipole_pattern():
    """p = 1 (N-type) carries -a_l: a small sphere radiates like an x-dipole."""
    assert mie_dipole_pattern_ratio() < 1e-4


@pytest.mark.parametrize("r", [0.08, 0.16, 0.24])
def test_mie_radius_derivative_fd(r):
    h = 1e-4
    d = mie.tmatrix_diag_dr(5, K0, r, 2.0)
    f = lambda rr: mie.tmatrix_diag(5, K0, rr, 2.0)
    fd = (-f(r + 2 * h) + 8 * f(r + h) - 8 * f(r - h) + f(r - 2 * h)) / (12 * h)
    assert np.max(np.abs(d - fd)) < 1e-8 * np.max(np.abs(d))
