"""Incident-field expansion coefficients (App. II).

Plane wave (App. II-A, Eqs. integrand_p_0 / integrand_p_1, explicit forms):
for a plane wave A e^{i k.x} travelling along
    k^ = (sin b cos a, sin b sin a, cos b)   (b = beta, a = alpha)
with transverse polarisation A (A . k^ = 0), the expansion about the origin
    A e^{i k.x} = sum a_{lmp}(b, a) RPhi_{lmp}(k x)
has
    a_{lm0} = -4 i^l     e^{-i m a} / sqrt(2l(l+1)) [ i m pi_l^{|m|}(b) (b^.A) + tau_l^{|m|}(b) (a^.A) ]
    a_{lm1} = -4 i^{l+1} e^{-i m a} / sqrt(2l(l+1)) [ tau_l^{|m|}(b) (b^.A) - i m pi_l^{|m|}(b) (a^.A) ]
with b^ = (cos a cos b, sin a cos b, -sin b), a^ = (-sin a, cos a, 0).
Reading: the printed first equality has "4 i^m"; the explicit forms (i^l) are
used (they reproduce the plane wave pointwise, see the tests).
About a scatterer at x_j the coefficients gain the phase e^{i k.x_j}.
"""
import math

import numpy as np

from .specfun import legendre_norm


def direction(beta, alpha):
    return np.array([math.sin(beta) * math.cos(alpha), math.sin(beta) * math.sin(alpha), math.cos(beta)])


def beta_hat(beta, alpha):
    return np.array([math.cos(alpha) * math.cos(beta), math.sin(alpha) * math.cos(beta), -math.sin(beta)])


def alpha_hat(beta, alpha):
    return np.array([-math.sin(alpha), math.cos(alpha), 0.0])


def planewave_coeffs(nmax, beta, alpha, A):
    """a_{lmp}(beta, alpha) for polarisation vector A (complex 3-vector)."""
    A = np.asarray(A, dtype=np.complex128)
    P, pi, tau = legendre_norm(nmax, beta)
    bA = beta_hat(beta, alpha) @ A
    aA = alpha_hat(beta, alpha) @ A
    L = nmax * (nmax + 2)
    out = np.zeros(2 * L, dtype=np.complex128)
    for l in range(1, nmax + 1):
        c = 1.0 / math.sqrt(2.0 * l * (l + 1))
        il = 1j ** (l % 4)
        for m in range(-l, l + 1):
            am = abs(m)
            e = complex(math.cos(m * alpha), -math.sin(m * alpha))
            n = l * (l + 1) + m - 1
            out[n] = -4.0 * il * e * c * (1j * m * pi[l, am] * bA + tau[l, am] * aA)
            out[L + n] = -4.0 * il * 1j * e * c * (tau[l, am] * bA - 1j * m * pi[l, am] * aA)
    return out


def planewave_incident(nmax, k, pos, beta, alpha, A):
    """a0 for every scatterer: shape (N, P), a0_j = e^{i k.x_j} a(beta, alpha)."""
    pos = np.asarray(pos, dtype=np.float64)
    a = planewave_coeffs(nmax, beta, alpha, A)
    kvec = k * direction(beta, alpha)
    ph = np.exp(1j * (pos @ kvec))
    return ph[:, None] * a[None, :]


def planewave_field(k, beta, alpha, A, pts):
    """The plane wave itself, A e^{i k.x}, at points pts (M, 3)."""
    pts = np.asarray(pts, dtype=np.float64)
    kvec = k * direction(beta, alpha)
    return np.exp(1j * (pts @ kvec))[:, None] * np.asarray(A, dtype=np.complex128)[None, :]
