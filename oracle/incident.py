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


# ----------------------------------------------------------------------------
# Jinc sources (App. II, "Computation of jinc sources").
#
# Readings: the sampling kernel is the cylindrical J_1 (the Fourier form of the
# paper integrates to J_1(k0 rho)/(k0 rho), not to the spherical j_1), and a
# source on a grid of pitch a carries the weight of its cell, a^2/(4 pi^2), so that
# for a field band-limited to the disc |k^T| < k0 (and a small enough that no
# other reciprocal-lattice image of the band falls in the disc)
#     E^T(x^T, z0) = sum_s E^T(x_s, z0) (a^2 k0^2 / (2 pi)) J_1(k0 rho_s)/(k0 rho_s),
# i.e. each source is (a^2/(4 pi^2)) int_{|k^T|<k0} A_s e^{i k^T.(x^T - x_s)} d^2k^T.
# On the paper's lambda/2 grid (a = pi/k0) the kernel is (pi/2) J_1/(k0 rho) and the
# weight 1/(4 k0^2).
# Each plane-wave component is propagated with e^{i k_z (z - z0)} and completed
# to a transverse vector A(k^T) = A^T - z^ (k^T.A^T)/k_z. With k^T = k0 sin b
# (cos a, sin a), d^2k^T = k0^2 sin b cos b db da, the coefficients about a
# sphere at x_j of a group of sources are
#     a0_j = (a k0 / (2 pi))^2 int db da sin b cos b e^{i k.(x_j - z0 z^)} a_lmp(b, a; A(k^T)),
#     A(k^T) = S^T - z^ tan b (k^T^.S^T),   S^T(k^T) = sum_s A_s e^{-i k^T.x_s}.
# The quadrature rule is part of the definition: Gauss-Legendre in b on
# [0, pi/2] (n_beta nodes) times the trapezoid rule in a (n_alpha nodes).
# ----------------------------------------------------------------------------

def jinc_rule(n_beta, n_alpha):
    """Nodes and weights: (beta[nb], w_beta[nb], alpha[na], w_alpha)."""
    xg, wg = np.polynomial.legendre.leggauss(n_beta)
    beta = (xg + 1.0) * (math.pi / 4.0)  # map [-1, 1] -> [0, pi/2]
    wb = wg * (math.pi / 4.0)
    alpha = np.arange(n_alpha) * (2.0 * math.pi / n_alpha)
    return beta, wb, alpha, 2.0 * math.pi / n_alpha


def jinc_rule_size(k0, extent):
    """Rule that resolves phases up to k0 * extent (extent: the largest distance
    between a sphere and a source, transverse and along z combined)."""
    kd = k0 * extent
    n_beta = int(math.ceil(kd * math.pi / 4.0)) + 24
    n_alpha = int(math.ceil(kd)) + 32
    n_alpha += (-n_alpha) % 4
    return n_beta, n_alpha


def jinc_group_coeffs(nmax, k0, pos, src_xy, src_A, z0, rule, pitch=None):
    """a0 (N, P) of one group of jinc sources (positions src_xy (S, 2) on the plane
    z = z0, transverse amplitudes src_A (S, 2) complex) about every sphere; the
    sources lie on a grid of the given pitch (default lambda/2 = pi/k0)."""
    cell = ((pitch if pitch else math.pi / k0) * k0 / (2.0 * math.pi)) ** 2
    pos = np.asarray(pos, dtype=np.float64)
    src_xy = np.asarray(src_xy, dtype=np.float64)
    src_A = np.asarray(src_A, dtype=np.complex128)
    beta, wb, alpha, wa = rule
    L = nmax * (nmax + 2)
    out = np.zeros((pos.shape[0], 2 * L), dtype=np.complex128)
    for ib, b in enumerate(beta):
        sb, cb = math.sin(b), math.cos(b)
        for a in alpha:
            ca, sa = math.cos(a), math.sin(a)
            kx, ky, kz = k0 * sb * ca, k0 * sb * sa, k0 * cb
            # group spectrum S^T(k^T)
            ph = np.exp(-1j * (kx * src_xy[:, 0] + ky * src_xy[:, 1]))
            Sx = np.sum(src_A[:, 0] * ph)
            Sy = np.sum(src_A[:, 1] * ph)
            kdotS = ca * Sx + sa * Sy
            A = np.array([Sx, Sy, -math.tan(b) * kdotS])
            coef = planewave_coeffs(nmax, b, a, A)
            w = cell * wb[ib] * wa * sb * cb
            phase = np.exp(1j * (kx * pos[:, 0] + ky * pos[:, 1] + kz * (pos[:, 2] - z0)))
            out += (w * phase)[:, None] * coef[None, :]
    return out
